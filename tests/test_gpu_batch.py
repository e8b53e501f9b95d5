"""Batched form: every instance of a mixed-N batch against its own oracle run."""
import numpy as np
import pytest

from oracle import system as SYS
from paper_1812_11626_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1812_11626_gb300 import gksl
    return gksl


@pytest.mark.parametrize("tile", ["auto", "0", "1", "3", "p1", "p3"])
def test_batch_mixed_n_vs_oracle(G, tile, monkeypatch):
    """Mixed N in one batch, every instance path: the autotuner's choice, the 16-byte-gather path
    (tile 0), the scalar paths on rows with 1 and 3 instances per lane, and the same on pair units
    (p1, p3: the S and J rows of a pair read one merged column list), each against per-instance
    oracle runs."""
    if tile != "auto":
        monkeypatch.setenv("GKSL_BATCH_TILE", tile)
    sizes = [(5, 3), (9, 40), (12, 70)]   # (N, instances): chunk widths 1..3 warps of lanes
    rng = np.random.default_rng(3)
    ctxs, A, g, inst = [], [], [], []
    for N, B in sizes:
        d = W.dimer(N)
        d.rate = 1.0 / (N - 1)   # group rate gamma = 1 per boson; g_b = gamma_b scales it
        ctxs.append(G.dimer_context(d))
        for _ in range(B):
            a, gam = 0.5 + 2.5 * rng.random(), 10 ** (-2 + 2 * rng.random())
            A.append(a)
            g.append(gam)
            inst.append((N, a, gam))
    b = G.gksl_batch_create(ctxs, [B for _, B in sizes], A, g)
    try:
        spp, periods = 3000, 2   # above the RK4 stability bound of every instance
        G.gksl_batch_propagate(b, [spp] * len(sizes), [spp * periods] * len(sizes), spp)
        for i in list(range(0, len(inst), 7)) + [len(inst) - 1]:
            N, a, gam = inst[i]
            d = W.dimer(N, dict(A=a, gamma=gam))
            u = SYS.unfold_dimer(d)
            v_ref, _ = SYS.propagate_dimer(d, u, spp, spp * periods)
            v = np.zeros(N * N - 1)
            G.gksl_batch_get_state(b, i, v)
            assert np.abs(v - v_ref).max() < 1e-5, (i, N, np.abs(v - v_ref).max())
        for gi in range(len(sizes)):
            ipl, us = G.gksl_batch_info(b, gi)
            if tile == "auto":
                assert 1 <= ipl <= 4 and us > 0
            else:   # forced: no timing, the forced width (4 for the 16-byte path)
                assert ipl == (4 if tile == "0" else int(tile.lstrip("p"))) and us == 0
                path = G.gksl_batch_group_stats(b, gi)[4]
                assert path == (2 if tile.startswith("p") else (0 if tile == "0" else 1))
    finally:
        G.gksl_batch_destroy(b)
        for c in ctxs:
            G.gksl_destroy(c)


def test_batch_256_seeded_instances_sampled(G, record):
    """The batched workload at full size (256 seeded instances, N in {50, 100, 200}) in the launch
    configuration the benchmark times: a tenth of a period per group at its stable step size;
    three instances of every group against their own oracle runs (FP32 bulk tolerance)."""
    inst = W.batch_instances(256, 1812)
    b, ctxs, groups = G.dimer_batch(inst)
    try:
        spps = [spp for _, _, spp in groups]
        steps = [max(1, s // 10) for s in spps]
        G.gksl_batch_propagate(b, spps, steps, 0)
        pos, worst = 0, 0.0
        for (N, idx, spp), n in zip(groups, steps):
            for j in (0, len(idx) // 2, len(idx) - 1):
                x = inst[idx[j]]
                d = W.dimer(N, dict(A=x["A"], gamma=x["gamma"]))
                u = SYS.unfold_dimer(d)
                v_ref, _ = SYS.propagate_dimer(d, u, spp, n)
                v = np.zeros(N * N - 1)
                G.gksl_batch_get_state(b, pos + j, v)
                worst = max(worst, np.abs(v - v_ref).max())
                assert np.abs(v - v_ref).max() < 1e-5, (N, j, np.abs(v - v_ref).max())
            pos += len(idx)
        record("max_abs_dv_vs_oracle_9_sampled_instances", worst)
    finally:
        G.gksl_batch_destroy(b)
        for c in ctxs:
            G.gksl_destroy(c)


@pytest.mark.parametrize("tile", ["auto", "0", "2", "p2"])
def test_bifurcation_scan_vs_oracle(G, tile, monkeypatch):
    """U-scan of the dimer as one batch (a per-instance interaction weight): populations
    diag rho after 2 periods for 8 values of U against single-instance oracle runs, and the
    populations are a probability distribution; with the scanned component as the fourth value
    channel of the 16-byte path (tile 0), the scalar row path (2) and the pair path (p2)."""
    if tile != "auto":
        monkeypatch.setenv("GKSL_BATCH_TILE", tile)
    N = 12
    U = np.linspace(0.0, 1.4, 8)
    pops, spp, res, per = G.bifurcation_scan(N, U, transient=1, max_periods=1)
    assert per == 2 and np.all(np.isfinite(res)) and res.max() > 0
    from oracle import basis as OB
    for i in (0, 3, 7):
        d = W.dimer(N, dict(U=float(U[i])))
        u = SYS.unfold_dimer(d)
        v_ref, _ = SYS.propagate_dimer(d, u, spp, 2 * spp)
        ref = np.real(np.diag(OB.rho_from_v(v_ref, N=N)))
        assert np.abs(pops[i] - ref).max() < 1e-5, (i, np.abs(pops[i] - ref).max())
    assert np.abs(pops.sum(1) - 1).max() < 1e-12 and pops.min() > -1e-6


def test_batch_fp64_correction_only_matches_fp64(G):
    """With an FP64 step every step the batch reproduces the FP64 single-instance path."""
    d = W.dimer(7)
    ctx = G.dimer_context(d)
    try:
        b = G.gksl_batch_create([ctx], [2], [d.params["A"], 0.3], [1.0, 0.5])
        try:
            G.gksl_batch_propagate(b, [400], [400], 1)
            u = SYS.unfold_dimer(d)
            v_ref, _ = SYS.propagate_dimer(d, u, 400, 400)
            v = np.zeros(48)
            G.gksl_batch_get_state(b, 0, v)
            assert np.abs(v - v_ref).max() < 1e-10
        finally:
            G.gksl_batch_destroy(b)
    finally:
        G.gksl_destroy(ctx)


def test_asymptotic_state_converges_vs_oracle(G, record):
    """Floquet asymptotic state (Sec. I, Sec. V): N = 20, eight interactions U, FP64 throughout;
    after the transient of 10 periods the batch runs period by period until every instance's
    period-map residual max |v(kT) - v((k-1)T)| <= 1e-8.  The residuals and the populations at the
    final period end match the oracle's RK4 run for the same number of periods (its residual taken
    from its own period-end states)."""
    from oracle import basis as OB
    from oracle import propagate as OP
    N = 20
    U = np.linspace(0.1, 1.0, 8)
    pops, spp, res, per = G.bifurcation_scan(N, U, transient=10, tol=1e-8, max_periods=80, correction_every=1)
    record("periods_to_1e-8", per)
    assert np.all(res <= 1e-8) and 10 < per < 90, (per, res.max())
    for i in (0, 4, 7):
        d = W.dimer(N, dict(U=float(U[i])))
        u = SYS.unfold_dimer(d)
        _, outs = SYS.propagate_dimer(d, u, spp, per * spp, emit_every=spp, threaded=True)
        r_ref = np.abs(outs[-1] - outs[-2]).max()
        ref = np.real(np.diag(OB.rho_from_v(outs[-1], N=N)))
        assert np.abs(pops[i] - ref).max() < 1e-10, (i, np.abs(pops[i] - ref).max())
        assert abs(res[i] - r_ref) <= 1e-12 + 1e-6 * r_ref, (i, res[i], r_ref)


def test_bifurcation_scan_n100_32_values_vs_oracle(G, record):
    """The bifurcation diagram at size: N = 100 (D = 9 999), 32 interactions U in [0.05, 1], one
    batch, FP32 bulk with an FP64 step per period, the paper's transient of 10 periods and one
    more period for the residual; populations and the state of three sampled U values against the
    oracle's FP64 RK4 (FP32 tolerances: 1e-5 on v, 1e-4 on populations)."""
    import time
    from oracle import basis as OB
    N = 100
    U = np.linspace(0.05, 1.0, 32)
    t0 = time.perf_counter()
    pops, spp, res, per = G.bifurcation_scan(N, U, transient=10, max_periods=1)
    sec = time.perf_counter() - t0
    record("steps_per_period", spp)
    record("instance_steps_per_s_incl_assembly", 32 * per * spp / sec)
    record("max_period_residual", res.max())
    assert per == 11 and np.all(np.isfinite(res))
    assert np.abs(pops.sum(1) - 1).max() < 1e-10 and pops.min() > -1e-6
    worst = 0.0
    for i in (0, 15, 31):
        d = W.dimer(N, dict(U=float(U[i])))
        u = SYS.unfold_dimer(d)
        v_ref, _ = SYS.propagate_dimer(d, u, spp, per * spp, threaded=True)
        ref = OB.populations_from_v(v_ref, N)
        worst = max(worst, np.abs(pops[i] - ref).max())
        assert np.abs(pops[i] - ref).max() < 1e-4, (i, np.abs(pops[i] - ref).max())
    record("max_abs_population_diff_vs_oracle", worst)
