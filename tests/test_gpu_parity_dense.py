"""Full-size parity from a dense state: every row of the unfolded system gathers live data.

Starting from the benchmark's pure state |0, M><0, M| most rows of Q0 + eps Q1 multiply zeros for
the first steps (at N = 1000 nine rows in ten), so a wrong column or offset there would pass.
Here the initial state is a seeded rank-3 density matrix (``workloads.random_density_matrix``):
every entry of rho is nonzero, so is every component of v(0) (Eq. 6), and every row of the first
stage derivative k1 = (Q0 + E Q1) v(0) + K is checked to be nonzero in at least 99 % of the rows
before any comparison.  The GPU sets v(0) from rho with its own expansion (gksl_set_rho0); the
oracle expands rho by the entry formulas of the generator basis (``basis.expand_dense``), unfolds
the dimer by the definition Tr(F_s L(F_m)) and runs classical RK4 (Sec. IV step 3.1) on its own
matrices (``native.rk4``, the same map as ``propagate.rk4`` on all host cores).

Tolerances, stated per precision: FP64 1e-10 absolute on v (|v| <= 1) and 1e-9 of the largest
change of any component over the run; FP32 bulk form 1e-5 absolute on v and 1e-4 of that change.
Runs of 70 steps span one 64-step CUDA graph and a remainder.
"""
import os

import numpy as np
import pytest

from oracle import basis as OB
from oracle import system as SYS
from paper_1812_11626_gb300 import workloads as W

pytestmark = pytest.mark.gpu
TOL64, REL64 = 1e-10, 1e-9
TOL32, REL32 = 1e-5, 1e-4
NSTEPS = 70
SEED = 1812


@pytest.fixture(scope="module")
def G():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1812_11626_gb300 import gksl
    return gksl


class _Case:
    """Oracle side of one dimer size: matrices, v(0) of the dense state and the reference run."""

    def __init__(self, N, nsteps=NSTEPS):
        self.d = W.dimer(N)
        self.N, self.D = N, N * N - 1
        self.re, self.im = W.random_density_matrix(N, 3, SEED + N)
        self.v0 = OB.expand_dense(self.re + 1j * self.im).real
        self.u = SYS.unfold_dimer(self.d)
        p = self.d.params
        Q0 = self.u.q0(p["J"], p["U"], self.d.rate)
        k1 = Q0 @ self.v0 + p["E"] * (self.u.Q1 @ self.v0) + self.d.rate * self.u.K1
        self.live_rows = float(np.mean(np.abs(k1) > 1e-14 * np.abs(k1).max()))
        self.nsteps = nsteps
        self.ref = {}

    def reference(self, spp):
        if spp not in self.ref:
            self.ref[spp], _ = SYS.propagate_dimer(self.d, self.u, spp, self.nsteps, v0=self.v0, threaded=True)
        return self.ref[spp]

    def errors(self, v, spp):
        ref = self.reference(spp)
        err = np.abs(v - ref).max()
        change = np.abs(ref - self.v0).max()
        return err, err / change


def _run(G, ctx, case, spp, precision, env=None):
    """Set v(0) from the dense rho on the GPU, run case.nsteps steps with the stage-kernel choice
    given by `env` (GKSL_RK4_VARIANT / GKSL_RK4_COLUMNS), return (v, info)."""
    env = env or {}
    old = {k: os.environ.get(k) for k in ("GKSL_RK4_VARIANT", "GKSL_RK4_COLUMNS")}
    for k in old:
        os.environ.pop(k, None)
    os.environ.update(env)
    try:
        G.gksl_assemble(ctx, G.GKSL_ASM_FP32)   # a fresh assembly chooses the stage kernel again
        G.gksl_set_rho0(ctx, case.re, case.im)
        out = np.zeros((1, case.D))
        G.gksl_propagate(ctx, spp, case.nsteps, precision, 0, case.nsteps, out)
        return out[0], G.gksl_get_info(ctx)
    finally:
        for k, v in old.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


@pytest.fixture(scope="module")
def n1000(G):
    case = _Case(1000)
    ctx = G.dimer_context(case.d, flags=G.GKSL_ASM_FP32)
    yield G, ctx, case
    G.gksl_destroy(ctx)


N1000_FP64 = [
    ("v0_32bit", {"GKSL_RK4_VARIANT": "0", "GKSL_RK4_COLUMNS": "32"}, 0, 0),
    ("v0_16bit", {"GKSL_RK4_VARIANT": "0"}, 0, 1),
    ("pdl_16bit", {"GKSL_RK4_VARIANT": "3"}, 3, 1),
    ("timer_choice", {}, None, None),
]


@pytest.mark.parametrize("name,env,variant,c16", N1000_FP64, ids=[c[0] for c in N1000_FP64])
def test_n1000_fp64_dense_state(n1000, record, name, env, variant, c16):
    """N = 1000 (D = 999 999) FP64 at the stable step size: variant 0 with 32-bit columns (the
    benchmark's kernel), variant 0 and pdl with 16-bit columns (escaped rows included), and the
    variant the timer picks unforced, each element by element against the oracle."""
    G, ctx, case = n1000
    assert case.live_rows >= 0.99, case.live_rows
    spp = G.gksl_min_stable_steps(ctx)
    v, info = _run(G, ctx, case, spp, 64, env)
    if variant is not None:
        assert info.rk4_variant[0] == variant and info.rk4_compact[0] == c16
    if c16:
        assert info.compact_escaped_rows > 0
    err, rel = case.errors(v, spp)
    record("live_row_fraction", case.live_rows)
    record("max_abs_dv_vs_oracle", err)
    record("rel_to_max_change", rel)
    assert err < TOL64 and rel < REL64, (err, rel)


def test_n1000_fp32_dense_state(n1000, record):
    """N = 1000 FP32 bulk form with the 16-bit columns and their escaped rows (the timer's choice at
    this size), and with the 32-bit columns forced, against the oracle's FP64 RK4."""
    G, ctx, case = n1000
    spp = G.gksl_min_stable_steps(ctx)
    for name, env, c16 in (("c16", {"GKSL_RK4_VARIANT": "0"}, 1),
                           ("c32", {"GKSL_RK4_VARIANT": "0", "GKSL_RK4_COLUMNS": "32"}, 0)):
        v, info = _run(G, ctx, case, spp, 32, env)
        assert info.rk4_compact[1] == c16
        err, rel = case.errors(v, spp)
        record(f"{name}_max_abs_dv_vs_oracle", err)
        record(f"{name}_rel_to_max_change", rel)
        assert err < TOL32 and rel < REL32, (name, err, rel)


@pytest.fixture(scope="module")
def n300():
    return _Case(300)


@pytest.mark.parametrize("variant", ["0", "1", "2", "3"])
def test_n300_every_variant_dense_state(G, n300, record, variant):
    """N = 300 (D = 89 999): each of the four stage-kernel variants in both precisions from the
    dense state against the oracle."""
    case = n300
    assert case.live_rows >= 0.99, case.live_rows
    ctx = G.dimer_context(case.d, flags=G.GKSL_ASM_FP32)
    try:
        spp = G.gksl_min_stable_steps(ctx)
        for prec, tol, rtol in ((64, TOL64, REL64), (32, TOL32, REL32)):
            v, info = _run(G, ctx, case, spp, prec, {"GKSL_RK4_VARIANT": variant})
            assert info.rk4_variant[0 if prec == 64 else 1] == int(variant)
            err, rel = case.errors(v, spp)
            record(f"fp{prec}_max_abs_dv_vs_oracle", err)
            record(f"fp{prec}_rel_to_max_change", rel)
            assert err < tol and rel < rtol, (prec, err, rel)
    finally:
        G.gksl_destroy(ctx)

