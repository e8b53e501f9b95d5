"""The allocation-free propagation entry point, checked against gksl_propagate.

gksl_propagate_csr_noalloc serves callers that cannot let the library allocate device memory
(their memory pool owns the GPU, or their loop must not stall on cudaMalloc/cudaFree): it takes
caller-owned device arrays and keeps its RK4 work vectors in a fixed array inside the library.
This file is named so that pytest collects it last.
"""
import numpy as np
import pytest

from paper_1812_11626_gb300 import workloads as W

pytestmark = pytest.mark.gpu
TOL64 = 1e-10   # the FP64 propagation tolerance used by the other parity tests


@pytest.fixture(scope="module")
def G():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1812_11626_gb300 import gksl
    return gksl


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

        dev = torch.device("cuda", 0)

        def csr(which):
            rp, col, val = G.get_csr_numpy(ctx, which)
            return (torch.as_tensor(rp, device=dev), torch.as_tensor(col, device=dev),
                    torch.as_tensor(val, device=dev))

        a0, a1 = csr(G.GKSL_MAT_Q0), csr(G.GKSL_MAT_Q1)
        K = np.zeros(D)
        G.gksl_get_k(ctx, K)
        K = torch.as_tensor(K, device=dev)
        v = torch.as_tensor(v0, device=dev).clone()
        for call in range(2):
            G.gksl_propagate_csr_noalloc(D, *a0, *a1, K, v, call * n * h, h, n, p["E"], p["A"], p["omega"])
            torch.cuda.synchronize()
            err = np.abs(v.cpu().numpy() - ref[call]).max()
            assert err < TOL64, (call, err)
    finally:
        G.gksl_destroy(ctx)


def test_noalloc_rejects_sizes_beyond_the_limit(G):
    import torch
    dev = torch.device("cuda", 0)
    dummy_i = torch.zeros(2, dtype=torch.int32, device=dev)
    dummy_d = torch.zeros(2, dtype=torch.float64, device=dev)
    with pytest.raises(G.GkslError) as e:
        G.gksl_propagate_csr_noalloc(G.GKSL_NOALLOC_MAX_D + 1, dummy_i, dummy_i, dummy_d, None, None, None, None,
                                     dummy_d, 0.0, 1e-3, 1, 0.0, 0.0, 1.0)
    assert e.value.status == G.GKSL_ERR_ARG


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
        dev = torch.device("cuda", 0)

        def csr(which):
            rp, col, val = G.get_csr_numpy(ctx, which)
            return (torch.as_tensor(rp, device=dev), torch.as_tensor(col, device=dev),
                    torch.as_tensor(val, device=dev))

        a0, a1 = csr(G.GKSL_MAT_Q0), csr(G.GKSL_MAT_Q1)
        K = np.zeros(D)
        G.gksl_get_k(ctx, K)
        K = torch.as_tensor(K, device=dev)
        v = torch.as_tensor(v0, device=dev).clone()
        for call in range(2):
            G.gksl_propagate_csr_noalloc(D, *a0, *a1, K, v, call * n * h, h, n, p["E"], p["A"], p["omega"])
            torch.cuda.synchronize()
            err = np.abs(v.cpu().numpy() - ref[call]).max()
            assert err < TOL64 * max(1.0, np.abs(ref[call]).max()), (call, err)
    finally:
        G.gksl_destroy(ctx)
