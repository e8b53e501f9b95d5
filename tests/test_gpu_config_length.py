"""Parity of the benchmark workloads at their stated lengths against the oracle.

* plain vs FP32-bulk dimer, N = 100 (D = 9 999): 100 periods at the stable 4 000 steps per
  period (the stated 2 000 diverge under RK4; the step count is raised, the length kept), FP64
  and FP32 bulk (one FP64 step per period) against the oracle's FP64 RK4 at every period end;
* batched, 256 seeded instances (N in {50, 100, 200}): one full period of every group at its
  stable step count, three instances per group against their own oracle runs;
* adjoint: the oracle's discrete-adjoint gradient (propagate.timeavg_adjoint) of the period mean
  of <n1 - n2> at N = 50 over period 2, FP64 and FP32.

Tolerances are the benchmark's: FP64 1e-10 absolute on v; FP32 1e-5 on v and 1e-4 on <n1 - n2>;
adjoint FP64 1e-9 and FP32 1e-5 of the gradient's largest component.  The long oracle runs use
the threaded C RK4 (the same map as the Python one, pinned alongside it).
"""
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


def test_n100_100_periods_fp64_and_fp32_vs_oracle(G, record):
    d = W.dimer(100)
    D = d.N * d.N - 1
    spp, periods = 4000, 100
    ctx = G.dimer_context(d)
    try:
        assert G.gksl_min_stable_steps(ctx) <= spp
        v64 = np.zeros((periods, D))
        G.gksl_propagate(ctx, spp, spp * periods, 64, 0, spp, v64)
        G.gksl_set_rho0(ctx, d.rho0_dense().real.copy())
        v32 = np.zeros((periods, D))
        G.gksl_propagate(ctx, spp, spp * periods, 32, spp, spp, v32)
    finally:
        G.gksl_destroy(ctx)
    u = SYS.unfold_dimer(d)
    _, ref = SYS.propagate_dimer(d, u, spp, spp * periods, emit_every=spp, threaded=True)
    ref = np.array(ref)
    w, c0 = OP.observable_weights(d.obs_diag)
    e64 = np.abs(v64 - ref).max()
    e32 = np.abs(v32 - ref).max(axis=1)
    o32 = np.abs((v32 - ref) @ w)
    record("fp64_max_abs_dv_vs_oracle_100_period_ends", e64)
    record("fp32_max_abs_dv_vs_oracle_100_period_ends", e32.max())
    record("fp32_obs_max_abs_diff_vs_oracle_100_period_ends", o32.max())
    record("fp32_obs_max_rel_to_M_vs_oracle", o32.max() / (d.N - 1))
    assert e64 < 1e-10, e64
    assert e32.max() < 1e-5, (int(e32.argmax()), e32.max())
    assert o32.max() < 1e-4, (int(o32.argmax()), o32.max())


def test_batch_256_one_full_period_per_group_vs_oracle(G, record):
    inst = W.batch_instances(256, 1812)
    b, ctxs, groups = G.dimer_batch(inst)
    try:
        spps = [spp for _, _, spp in groups]
        G.gksl_batch_propagate(b, spps, spps, min(spps))   # an FP64 step every min(spp) steps
        pos, worst_v, worst_o = 0, 0.0, 0.0
        for N, idx, spp in groups:
            for j in (0, len(idx) // 2, len(idx) - 1):
                x = inst[idx[j]]
                d = W.dimer(N, dict(A=x["A"], gamma=x["gamma"]))
                u = SYS.unfold_dimer(d)
                v_ref, _ = SYS.propagate_dimer(d, u, spp, spp, threaded=True)
                v = np.zeros(N * N - 1)
                G.gksl_batch_get_state(b, pos + j, v)
                w, _ = OP.observable_weights(d.obs_diag)
                ev, eo = np.abs(v - v_ref).max(), abs((v - v_ref) @ w)
                worst_v, worst_o = max(worst_v, ev), max(worst_o, eo)
                assert ev < 1e-5 and eo < 1e-4, (N, j, ev, eo)
            pos += len(idx)
        record("max_abs_dv_vs_oracle_9_instances_one_period", worst_v)
        record("max_abs_dobs_vs_oracle_9_instances_one_period", worst_o)
    finally:
        G.gksl_batch_destroy(b)
        for c in ctxs:
            G.gksl_destroy(c)


@pytest.fixture(scope="module")
def n50_oracle_gradient(G):
    d = W.dimer(50)
    ctx = G.dimer_context(d)
    try:
        S = G.gksl_min_stable_steps(ctx)
    finally:
        G.gksl_destroy(ctx)
    period = 2
    u = SYS.unfold_dimer(d)
    p = d.params
    h = 2 * np.pi / p["omega"] / S
    w, c0 = OP.observable_weights(d.obs_diag)
    sinw = lambda t: np.sin(p["omega"] * t)
    L, g = OP.timeavg_adjoint(u.q0(p["J"], p["U"], d.rate), u.Q1, d.rate * u.K1,
                              OP.eps_fn(p["E"], p["A"], p["omega"]), SYS.initial_v(d), w, c0, h, S, period,
                              dQ0=[None, u.R1, u.QJ, u.QU], dQ1=[(u.Q1, sinw), None, None, None],
                              dK=[None, u.K1, None, None])
    return d, S, period, L, g


@pytest.mark.parametrize("form", ["auto", "rows", "wide"])
@pytest.mark.parametrize("precision,tol", [(64, 1e-9), (32, 1e-5)])
def test_adjoint_n50_two_periods_vs_oracle_gradient(G, n50_oracle_gradient, precision, tol, record, form,
                                                    monkeypatch):
    # reverse-stage forms: the library's choice, channel by channel, and all of a row's stacked
    # slots loaded at once in both precisions
    env = {"auto": {}, "rows": {"GKSL_ADJ_WIDE": "0", "GKSL_ADJ_PIPE": "0"}, "wide": {"GKSL_ADJ_WIDE": "1"}}
    for k, v in env[form].items():
        monkeypatch.setenv(k, v)
    d, S, period, L, g = n50_oracle_gradient
    ctx = G.dimer_context(d)
    try:
        grad = np.zeros(4)
        loss = G.gksl_adjoint_timeavg(ctx, d.obs_diag, S, period, precision, grad)
    finally:
        G.gksl_destroy(ctx)
    rel = np.abs(grad - g).max() / np.abs(g).max()
    record("steps_per_period", S)
    record("loss_abs_diff_vs_oracle", abs(loss - L))
    record("grad_max_abs_diff_vs_oracle_over_max", rel)
    assert abs(loss - L) < (1e-11 if precision == 64 else 1e-5) * max(1.0, abs(L))
    assert rel < tol, (grad, g)
