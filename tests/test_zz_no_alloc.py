"""The allocation-free propagation entry point, checked against gksl_propagate and the oracle.

gksl_propagate_csr_noalloc serves callers that cannot let the library allocate device memory
(their memory pool owns the GPU, or their loop must not stall on cudaMalloc/cudaFree): it takes
caller-owned device arrays and keeps its RK4 work vectors in a fixed array inside the library.
This file is named so that pytest collects it last.
"""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import basis as OB
from oracle import native
from oracle import system as SYS
from paper_1812_11626_gb300 import workloads as W

pytestmark = pytest.mark.gpu
TOL64 = 1e-10   # the FP64 propagation tolerance used by the other parity tests


@pytest.fixture(scope="module")
def G():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1812_11626_gb300 import gksl
    return gksl


def _dev():
    import torch
    return torch.device("cuda", 0)


def _csr_tensors(X):
    """A scipy matrix as the (rowptr, col, val) device tensors the entry point takes."""
    import torch
    X = sp.csr_matrix(X)
    X.sort_indices()
    return (torch.as_tensor(X.indptr.astype(np.int32), device=_dev()),
            torch.as_tensor(X.indices.astype(np.int32), device=_dev()),
            torch.as_tensor(X.data.astype(np.float64), device=_dev()))


def _ctx_csr(G, ctx, which):
    import torch
    rp, col, val = G.get_csr_numpy(ctx, which)
    return (torch.as_tensor(rp, device=_dev()), torch.as_tensor(col, device=_dev()), torch.as_tensor(val, device=_dev()))


def test_noalloc_matches_propagate_on_two_calls(G):
    import torch
    d = W.dimer(20)
    ctx = G.dimer_context(d)
    try:
        D = d.N * d.N - 1
        p = d.params
        spp, n = 400, 150
        h = 2 * np.pi / p["omega"] / spp
        v0 = np.zeros(D)
        G.gksl_get_state(ctx, v0)
        ref = np.zeros((2, D))
        G.gksl_propagate(ctx, spp, 2 * n, 64, 0, n, ref)
        a0, a1 = _ctx_csr(G, ctx, G.GKSL_MAT_Q0), _ctx_csr(G, ctx, G.GKSL_MAT_Q1)
        K = np.zeros(D)
        G.gksl_get_k(ctx, K)
        K = torch.as_tensor(K, device=_dev())
        v = torch.as_tensor(v0, device=_dev()).clone()
        for call in range(2):
            G.gksl_propagate_csr_noalloc(D, *a0, *a1, K, v, call * n * h, h, n, p["E"], p["A"], p["omega"])
            torch.cuda.synchronize()
            err = np.abs(v.cpu().numpy() - ref[call]).max()
            assert err < TOL64, (call, err)
    finally:
        G.gksl_destroy(ctx)


@pytest.mark.parametrize("with_a1", [True, False])
@pytest.mark.parametrize("with_k", [True, False])
def test_noalloc_optional_a1_and_k_vs_oracle(G, with_a1, with_k):
    """The documented branches: A1 given or NULL (all three pointers) and K given or NULL, each
    against the oracle's RK4 of the same system (the N = 12 dimer's matrices by definition, from a
    dense state), on two calls in a row."""
    import torch
    d = W.dimer(12)
    u = SYS.unfold_dimer(d)
    p = d.params
    D = d.N * d.N - 1
    Q0 = u.q0(p["J"], p["U"], d.rate)
    Q1 = u.Q1 if with_a1 else None
    K = d.rate * u.K1 if with_k else None
    re, im = W.random_density_matrix(d.N, 3, 12)
    v0 = OB.expand_dense(re + 1j * im).real
    spp, n = 600, 100
    h = 2 * np.pi / p["omega"] / spp
    _, ref = native.rk4(Q0, Q1, K, p["E"], p["A"], p["omega"], v0, h, 2 * n, emit_every=n)
    a1 = _csr_tensors(Q1) if with_a1 else (None, None, None)
    Kt = torch.as_tensor(K, device=_dev()) if with_k else None
    v = torch.as_tensor(v0, device=_dev()).clone()
    for call in range(2):
        G.gksl_propagate_csr_noalloc(D, *_csr_tensors(Q0), *a1, Kt, v, call * n * h, h, n, p["E"], p["A"], p["omega"])
        torch.cuda.synchronize()
        err = np.abs(v.cpu().numpy() - ref[call]).max()
        assert err < TOL64, (call, err)


def test_noalloc_zero_steps_side_stream_and_no_allocation(G):
    """n_steps = 0 leaves v as it was; a call made inside a torch side-stream context runs on that
    stream, after the work that filled v there; and after a first call the entry point takes no
    device memory (cudaMemGetInfo's free bytes are the same before and after a second call)."""
    import torch
    d = W.dimer(16)
    u = SYS.unfold_dimer(d)
    p = d.params
    D = d.N * d.N - 1
    Q0 = u.q0(p["J"], p["U"], d.rate)
    a0, a1 = _csr_tensors(Q0), _csr_tensors(u.Q1)
    K = torch.as_tensor(d.rate * u.K1, device=_dev())
    re, im = W.random_density_matrix(d.N, 3, 16)
    v0 = OB.expand_dense(re + 1j * im).real
    spp, n = 800, 120
    h = 2 * np.pi / p["omega"] / spp
    v = torch.as_tensor(v0, device=_dev()).clone()
    G.gksl_propagate_csr_noalloc(D, *a0, *a1, K, v, 0.0, h, 0, p["E"], p["A"], p["omega"])
    torch.cuda.synchronize()
    assert np.array_equal(v.cpu().numpy(), v0)
    ref, _ = native.rk4(Q0, u.Q1, d.rate * u.K1, p["E"], p["A"], p["omega"], v0, h, n)
    src = torch.as_tensor(v0, device=_dev())
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        v2 = torch.empty(D, dtype=torch.float64, device=_dev())
        torch.cuda._sleep(2_000_000)          # the copy below lands well after the call is enqueued
        v2.copy_(src)
        G.gksl_propagate_csr_noalloc(D, *a0, *a1, K, v2, 0.0, h, n, p["E"], p["A"], p["omega"])
    side.synchronize()
    assert np.abs(v2.cpu().numpy() - ref).max() < TOL64
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    G.gksl_propagate_csr_noalloc(D, *a0, *a1, K, v, 0.0, h, n, p["E"], p["A"], p["omega"])
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert np.abs(v.cpu().numpy() - ref).max() < TOL64


def test_noalloc_rejects_bad_arguments_before_launching(G):
    """Arguments the kernels would index out of bounds are rejected with GKSL_ERR_ARG before any
    launch: a size beyond the limit, an int64 rowptr, float32 values, a short rowptr, a short v, a
    partial A1 triple; v is left untouched."""
    import torch
    d = W.dimer(6)
    u = SYS.unfold_dimer(d)
    D = d.N * d.N - 1
    rp, col, val = _csr_tensors(u.q0(1.0, 0.5, 0.1))
    v = torch.ones(D, dtype=torch.float64, device=_dev())
    big = G.GKSL_NOALLOC_MAX_D + 1
    cases = {
        "too large": (big, rp, col, val, None, None, None, None, v),
        "int64 rowptr": (D, rp.long(), col, val, None, None, None, None, v),
        "float32 values": (D, rp, col, val.float(), None, None, None, None, v),
        "short rowptr": (D, rp[:-1].contiguous(), col, val, None, None, None, None, v),
        "short v": (D, rp, col, val, None, None, None, None, v[:-1]),
        "partial A1": (D, rp, col, val, rp, None, None, None, v),
        "short col": (D, rp, col[:-2].contiguous(), val[:-2].contiguous(), None, None, None, None, v),
    }
    for name, args in cases.items():
        with pytest.raises(G.GkslError) as e:
            G.gksl_propagate_csr_noalloc(*args, 0.0, 1e-3, 1, 0.0, 0.0, 1.0)
        assert e.value.status == G.GKSL_ERR_ARG, name
    torch.cuda.synchronize()
    assert bool((v == 1).all())


def test_noalloc_at_the_size_limit(G):
    """The largest dimer that fits the fixed work array (N = 512, D = 262 143 <= 262 144): two
    calls of a few steps each against gksl_propagate at the stable step size."""
    import torch
    d = W.dimer(512)
    ctx = G.dimer_context(d)
    try:
        D = d.N * d.N - 1
        assert D <= G.GKSL_NOALLOC_MAX_D
        p = d.params
        spp = G.gksl_min_stable_steps(ctx)
        h = 2 * np.pi / p["omega"] / spp
        n = 6
        v0 = np.zeros(D)
        G.gksl_get_state(ctx, v0)
        ref = np.zeros((2, D))
        G.gksl_propagate(ctx, spp, 2 * n, 64, 0, n, ref)
        a0, a1 = _ctx_csr(G, ctx, G.GKSL_MAT_Q0), _ctx_csr(G, ctx, G.GKSL_MAT_Q1)
        K = np.zeros(D)
        G.gksl_get_k(ctx, K)
        K = torch.as_tensor(K, device=_dev())
        v = torch.as_tensor(v0, device=_dev()).clone()
        for call in range(2):
            G.gksl_propagate_csr_noalloc(D, *a0, *a1, K, v, call * n * h, h, n, p["E"], p["A"], p["omega"])
            torch.cuda.synchronize()
            err = np.abs(v.cpu().numpy() - ref[call]).max()
            assert err < TOL64 * max(1.0, np.abs(ref[call]).max()), (call, err)
    finally:
        G.gksl_destroy(ctx)


def test_noalloc_at_the_size_limit_dense_state_vs_oracle(G, record):
    """N = 512 from a dense seeded state (every component of v(0) nonzero, at least 99 % of the rows
    of the first stage derivative nonzero) on the oracle's own matrices: two calls of 35 steps at
    the stable step size against the oracle's RK4, element by element."""
    import torch
    d = W.dimer(512)
    u = SYS.unfold_dimer(d)
    p = d.params
    D = d.N * d.N - 1
    Q0 = u.q0(p["J"], p["U"], d.rate)
    K = d.rate * u.K1
    re, im = W.random_density_matrix(d.N, 3, 512)
    v0 = OB.expand_dense(re + 1j * im).real
    k1 = Q0 @ v0 + p["E"] * (u.Q1 @ v0) + K
    live = float(np.mean(np.abs(k1) > 1e-14 * np.abs(k1).max()))
    assert np.abs(v0).min() > 0 and live >= 0.99, live
    ctx = G.dimer_context(d)
    try:
        spp = G.gksl_min_stable_steps(ctx)
    finally:
        G.gksl_destroy(ctx)
    h = 2 * np.pi / p["omega"] / spp
    n = 35
    _, ref = native.rk4(Q0, u.Q1, K, p["E"], p["A"], p["omega"], v0, h, 2 * n, emit_every=n)
    v = torch.as_tensor(v0, device=_dev()).clone()
    a0, a1, Kt = _csr_tensors(Q0), _csr_tensors(u.Q1), torch.as_tensor(K, device=_dev())
    for call in range(2):
        G.gksl_propagate_csr_noalloc(D, *a0, *a1, Kt, v, call * n * h, h, n, p["E"], p["A"], p["omega"])
        torch.cuda.synchronize()
        err = np.abs(v.cpu().numpy() - ref[call]).max()
        change = np.abs(ref[call] - v0).max()
        record(f"call{call}_max_abs_dv_vs_oracle", err)
        assert err < TOL64 and err < 1e-9 * change, (call, err, change)
